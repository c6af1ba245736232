/*
 * libpff -- C ABI of the GB300 matrix-free phase-field fracture operator.
 *
 * Method: "Matrix-free phase-field modeling of fracture in micromechanical
 * testing simulations of inelastic materials".  Peric-Dettmer rheology
 * (Hooke, Maxwell and perfectly plastic Prandtl branches on Hencky strains,
 * Sec. 2, Box 1) in series with a phase-field fracture element (Sec. 3),
 * monolithic 4-field residual and Jacobian evaluated matrix-free on
 * tensor-product Q_p hexahedra (Sec. 4), with the p-multigrid pieces
 * (matrix-free diagonal, Chebyshev-Jacobi smoothing, p-prolongation and
 * restriction) that the paper's solver uses (Sec. 5).
 *
 * Conventions
 *   - Units: mm, MPa, s.
 *   - Mesh: structured box of nx*ny*nz affine hexahedra of size hx*hy*hz, order
 *     p (P = p + 1 Gauss-Lobatto-Legendre nodes per direction), Q Gauss points
 *     per direction (Q = p_fine + 1 on every multigrid level).
 *     Node (I,J,K) has id I + nnx*(J + nny*K), nnx = p*nx + 1, nny = p*ny + 1.
 *     Element e = ex + nx*(ey + ny*ez); its local node (a,b,c) is node
 *     (p*ex + a, p*ey + b, p*ez + c).
 *   - Vectors: structure of arrays [4][N_n] (u_x, u_y, u_z, phi), FP64
 *     (PFF_F64) or FP32 (PFF_F32) as the call states.
 *   - Quadrature point q = e*Q^3 + i + Q*(j + Q*k) (Gauss points ascending).
 *   - History, structure of arrays [15][N_q] of FP64: words 0-5 C_in^-1 of the
 *     Maxwell branch, 6-11 C_in^-1 of the Prandtl branch (Voigt order 11, 22,
 *     33, 23, 13, 12), 12 accumulated plastic strain, 13 history field H,
 *     14 phase field at the last converged step (phi_n).
 *   - Flags, one uint8 per quadrature point: bit0 Prandtl branch yielded,
 *     bit1 history field active (psi+ > H_n), bit2 theta = ln J >= 0.
 *   - Dirichlet mask: uint8 [4][N_n], 1 = prescribed.
 *
 * Memory and streams
 *   Every array argument is a DEVICE pointer owned by the caller unless stated
 *   otherwise; handles own the device buffers they allocate (history, stored
 *   linearisation, work space) and free them in pff_destroy_*.  `stream` is a
 *   cudaStream_t passed as void*; calls are asynchronous on it.  Kernel-side
 *   failures (eigen sweeps not converged, det F <= 0, non-finite values) set a
 *   status word that pff_get_status reads back.
 *
 * Errors
 *   Every call returns PFF_OK (0) or a negative PFF_ERR_* code; the message of
 *   the last failing call on this thread is available from
 *   pff_last_error_message().  No exception crosses the ABI.
 */
#ifndef PFF_H
#define PFF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFF_OK 0
#define PFF_ERR_INVALID -1   /* bad argument or handle */
#define PFF_ERR_CUDA -2      /* CUDA runtime error (launch, copy, allocation) */
#define PFF_ERR_DEVICE -3    /* kernel status word set (see pff_get_status) */
#define PFF_ERR_UNSUPPORTED -4

/* kernel status bits returned by pff_get_status */
#define PFF_STATUS_EIGEN 1       /* Jacobi eigen sweeps hit their cap (20) */
#define PFF_STATUS_DETF 2        /* det F <= 0 at some quadrature point */
#define PFF_STATUS_NONFINITE 4   /* non-finite residual integrand */
#define PFF_STATUS_PHASE 8       /* phase id >= nphase (phase 0 used) */
#define PFF_STATUS_RETURN 16     /* hardening return map: local Newton hit its cap (50) */
#define PFF_STATUS_PIPE 32       /* FP32-arithmetic level action (PFF_F32 or PFF_F32_BF16 words): a wait for staged words gave up (result invalid) */

/* PFF_DF64: FP64 vectors, the Jacobian action's contractions carried in
 * double-float arithmetic (pairs of FP32 words on the FP32 pipes, error about
 * 2^-47 of the magnitudes per operation instead of 2^-53) and the stored
 * linearisation read from its hi/lo FP32 planes (pff_op_enable_df).  Accepted
 * by pff_jacobian_apply and pff_jacobian_transpose_apply only.
 * PFF_F32_BF16: FP32 vectors and arithmetic, the stored linearisation read as
 * BF16 words (8 significant bits, relative rounding error <= 2^-9 per word;
 * pff_op_enable_bf16): the p-multigrid level precision that halves the word
 * stream.  Accepted by the actions and pff_chebyshev_smooth(_noalloc);
 * pff_assemble_diagonal, pff_prolong and pff_restrict treat it as PFF_F32. */
typedef enum { PFF_F64 = 0, PFF_F32 = 1, PFF_DF64 = 2, PFF_F32_BF16 = 3 } pff_prec;

typedef struct pff_ctx pff_ctx;
typedef struct pff_basis pff_basis;
typedef struct pff_restr pff_restr;
typedef struct pff_op pff_op;
typedef struct pff_level pff_level;

/* Material and global parameters (Table 2; Sec. 3, 3.1).  phase_params holds
 * nphase rows of 12 doubles:
 *   Gc, l0, E_inf, nu_inf, hasMaxwell, E1, nu1, eta_d, hasPrandtl, E2, nu2, sigma0
 * (eta_d may be +inf).  at = 1 (AT1, c0 = 8/3) or 2 (AT2, c0 = 2); eta =
 * residual stiffness of g = (1 - phi)^2 + eta (Eq. degr-funct); zeta = damage
 * viscosity (Sec. 3.1); dt = time step; s_phi = phase-field residual scale
 * (Eq. damage-residual-scaling).  Host memory; copied. */
typedef struct {
  int nphase;
  const double* phase_params;
  int at;
  double eta;
  double zeta;
  double dt;
  double s_phi;
} pff_problem;

/* Affine box: nx*ny*nz elements of size hx*hy*hz. */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
} pff_box;

/* Text of the last failing call on this thread (thread-local; empty if none;
 * valid until the next failing call on the thread). */
const char* pff_last_error_message(void);
/* ABI version of this library (1). */
int pff_version(void);
/* Kernels this library has launched in this process so far (all devices and
 * host threads; counted on the host at each launch).  The difference across a
 * region of calls is the number of kernels those calls launched. */
int64_t pff_kernel_launches(void);

/* Context: parameters of the constitutive model (host data, copied). */
int pff_create_context(pff_ctx** ctx, const pff_problem* problem);
int pff_destroy_context(pff_ctx* ctx);
/* Time step of the next residual (Sec. 5 load stepping; adaptive cut-back
 * shortens it): sets dt and the Maxwell factor mu dt / eta_d of every phase.
 * dt > 0; applies to every operator built on ctx from its next call on. */
int pff_context_set_time_step(pff_ctx* ctx, double dt);
/* Strain hardening of phase `phase`'s Prandtl branch (Eq.
 * plasticity-strain-hardening-law): sigma_y(ep) = sigma0 + H_lin ep +
 * (sigma_inf - sigma0)(1 - exp(-beta ep)), ep the accumulated plastic strain
 * (history word 12), returned by the local Newton of Box 2 on the degraded
 * consistency condition g q_tr - 3 g mu dgam - sigma_y(ep_n + dgam) = 0.
 * Contexts start perfectly plastic (H_lin = 0, sigma_inf = sigma0).  Requires
 * H_lin >= 0, beta >= 0, sigma_inf >= sigma0 (non-decreasing sigma_y). */
int pff_context_set_hardening(pff_ctx* ctx, int phase, double H_lin, double sigma_inf, double beta);

/* Basis: GLL(p+1) nodes, Gauss(q) points and weights, 1D interpolation B[q][p+1]
 * and collocated derivative D[q][q] (Sec. 4, B_I and B_xi).  1 <= p, p+1 <= q <= 5.
 * pff_basis_get copies the 1D tables to host arrays (any may be NULL):
 * xg[p+1], xq[q], wq[q], B[q*(p+1)], Dc[q*q]. */
int pff_create_basis(pff_ctx* ctx, int p, int q, pff_basis** basis);
int pff_basis_get(const pff_basis* basis, double* xg, double* xq, double* wq, double* B, double* Dc);
int pff_destroy_basis(pff_basis* basis);

/* Element restriction E (Sec. 4): the structured box map, or explicit offsets
 * (device int32 [nel][(p+1)^3] of node ids, borrowed: must stay valid while
 * operators built on it are used).  nnodes = nodes per field. */
int pff_create_restriction(pff_ctx* ctx, const pff_box* box, int p, const int32_t* offsets_or_null,
                           int64_t nnodes, pff_restr** restr);
int pff_destroy_restriction(pff_restr* restr);

/* Fine-level operator: allocates the quadrature-point state (committed and
 * trial history, phase ids, flags), the FP64 stored linearisation
 * (70 words per point, 67 of them used on an affine box) and the residual
 * work space. */
int pff_create_operator(pff_ctx* ctx, pff_basis* fine, pff_restr* restr, pff_op** op);
int pff_destroy_operator(pff_op* op);
/* Also keep an FP32 copy of the stored linearisation (written by pff_residual),
 * needed by PFF_F32 applies.  Disabling frees it (and the PFF_DF64 planes). */
int pff_op_enable_f32(pff_op* op, int enable);
/* Keep the stored linearisation also as two FP32 planes hi = fl32(w),
 * lo = fl32(w - hi) (written by pff_residual; 8 more bytes per word than FP64
 * alone), needed by PFF_DF64 applies.  The hi plane doubles as the FP32 copy,
 * so enabling also enables FP32.  Disabling stops the lo updates and keeps the
 * memory until pff_op_enable_f32(op, 0). */
int pff_op_enable_df(pff_op* op, int enable);
/* Keep the stored linearisation also as BF16 words (72 per point, 144 bytes;
 * written by pff_residual, round to nearest even from FP64), needed by
 * PFF_F32_BF16 applies.  Disabling frees them. */
int pff_op_enable_bf16(pff_op* op, int enable);
/* Deterministic transposed contractions (race-free reruns): with enable = 1
 * the element kernels of pff_residual, the actions of every level of op (all
 * precisions, pff_jacobian_apply_host included), pff_assemble_diagonal and
 * pff_restrict leave their element values in a buffer ([nel][4][(p+1)^3] doubles, allocated
 * here), and one thread per node sums its incident elements' values in a
 * fixed order instead of the atomic scatter-add, so repeated calls give
 * bitwise identical results.  Calls on op must then not overlap on the GPU
 * (they share the buffer).  Needs the structured element numbering.  The
 * reaction and the adjoint keep the atomic scatter. */
int pff_op_set_deterministic(pff_op* op, int enable);
int64_t pff_op_num_qpoints(const pff_op* op);
int64_t pff_op_num_nodes(const pff_op* op);

/* Quadrature-point state: phase ids (uint8 [N_q]) and committed history
 * (FP64 [15][N_q]); device pointers, copied. */
int pff_set_qpoint_state(pff_op* op, const uint8_t* phase, const double* hist_committed, void* stream);
/* Dirichlet data of the fine level: mask uint8 [4][N_n] and values FP64
 * [4][N_n] (device, copied; values may be NULL = zero; mask NULL = none). */
int pff_set_dirichlet(pff_op* op, const uint8_t* mask, const double* values, void* stream);

/* Mapped mesh (curved or distorted hexahedra on the same logical grid and
 * restriction): X = nodal coordinates [3][N_n] (device, FP64, read once) of
 * the isoparametric element maps X(xi) = sum_a X_a N_a(xi).  Stores d xi / dX
 * and w_q det J at every Gauss point (10 FP64 words per point); from then on
 * the residual, the stored linearisation (all words in the parent frame, plus
 * three off-diagonal phase-gradient words) and every level operator use them.
 * X = NULL returns to the affine box of the restriction.  Fails with
 * PFF_ERR_INVALID (and keeps the box) if det J <= 0 at some Gauss point.
 * Synchronises the stream. */
int pff_op_set_geometry(pff_op* op, const double* X, void* stream);

/* Residual R(z) (Eq. matrix-free-residual-compact), FP64: r = internal
 * residual on free DoFs, r = z - ubar on Dirichlet DoFs.  Also writes the
 * trial history (Box 1 step 4), the flags, and the stored linearisation used
 * by every Jacobian action until the next call. */
int pff_residual(pff_op* op, const double* z, double* r, void* stream);

/* z = ubar on the Dirichlet DoFs set by pff_set_dirichlet (other entries kept). */
int pff_apply_dirichlet(pff_op* op, double* z, void* stream);
/* Reaction: sums, per field, of the internal force vector (Eq.
 * matrix-free-residual-compact without Dirichlet rows) over the DoFs selected
 * by sel (uint8 [4][N_n], device), for the state of the last pff_residual.
 * out4 is a HOST array of 4 doubles; synchronises the stream.  Allocates its
 * work vector on first use. */
int pff_reaction(pff_op* op, const uint8_t* sel, double* out4, void* stream);

/* Multigrid level built on the fine operator's quadrature points (coarse
 * Lagrange basis of order p_level evaluated at the fine Gauss points, sharing
 * the fine stored linearisation, i.e. the Galerkin operator P^T A P).
 * p_level = the fine order gives the fine operator itself. */
int pff_create_level(pff_op* fine, int p_level, pff_level** level);
int pff_destroy_level(pff_level* level);
int64_t pff_level_num_nodes(const pff_level* level);
/* Dirichlet mask of this level (uint8 [4][N_n(level)], device, copied; NULL = none).
 * The fine level created with p_level = fine order uses the operator's mask. */
int pff_level_set_mask(pff_level* level, const uint8_t* mask, void* stream);

/* Jacobian action y = J x (Eq. matrix-free-jacobian) with Dirichlet rows and
 * columns replaced by the identity: y = (I-M) J (I-M) x + M x.  x, y are
 * [4][N_n(level)] of the given precision. */
int pff_jacobian_apply(pff_level* level, pff_prec prec, const void* x, void* y, void* stream);
/* Transposed action y = J^T x (same Dirichlet treatment). */
int pff_jacobian_transpose_apply(pff_level* level, pff_prec prec, const void* x, void* y, void* stream);
/* The Jacobian action y = J x of pff_jacobian_apply with x and y in HOST
 * memory (4 N_n entries each, FP64 for PFF_F64 / PFF_DF64, FP32 for PFF_F32 /
 * PFF_F32_BF16; page-locked memory, e.g. cudaHostAlloc or cudaHostRegister,
 * lets the copies overlap the computation, pageable memory serialises them).
 * The element blocks run in `nchunks` chunks in element order (rounded to whole
 * waves of the element kernel); each chunk's node layers are uploaded ahead of
 * it on a second stream and the node layers no later chunk touches are
 * downloaded on a third while later chunks compute.  Asynchronous on
 * `stream`: x_host must stay unchanged and y_host unread until the stream has
 * passed this call.  The first call on a level allocates its device staging
 * (two vectors of 8 bytes per entry), two streams and four events, freed by
 * pff_destroy_level.  Needs the structured restriction (no explicit offsets). */
int pff_jacobian_apply_host(pff_level* level, pff_prec prec, const void* x_host, void* y_host, int nchunks,
                            void* stream);
/* Diagonal of J (1 on Dirichlet DoFs). */
int pff_assemble_diagonal(pff_level* level, pff_prec prec, void* diag, void* stream);

/* p-transfer between a coarse level and the next finer one (same element
 * grid): prolongation x_f = P x_c with P[f, c] = coarse Lagrange basis at the
 * fine GLL node, rows of fine Dirichlet DoFs and columns of coarse Dirichlet
 * DoFs removed; restriction r_c = P^T r_f. */
int pff_prolong(pff_level* coarse, pff_level* fine, pff_prec prec, const void* xc, void* xf, void* stream);
int pff_restrict(pff_level* coarse, pff_level* fine, pff_prec prec, const void* rf, void* rc, void* stream);

/* Chebyshev smoothing of J x = b preconditioned by diag (Saad, Alg. 12.1)
 * on the eigenvalue interval [lmin, lmax] of D^-1 J: `degree` Jacobian
 * actions; x updated in place.  work: 3 vectors [3][4][N_n] of the given
 * precision (caller-owned scratch). */
int pff_chebyshev_smooth(pff_level* level, pff_prec prec, int degree, double lmin, double lmax,
                         const void* diag, const void* b, void* x, void* work, void* stream);

/* The same smoother without caller-provided work space, for callers that may not
 * allocate device memory where they smooth (memory owned by another allocator or
 * a budget fixed at start-up; loops where cudaMalloc/cudaFree would synchronise
 * the device).  The paper has no counterpart: it is an interface convenience.
 * The three work vectors come from one array compiled into the library (up to
 * 4*N_n(level) = 2 097 152 entries per vector, 48 MiB, held by every GPU that
 * loads the library until exit); larger levels are rejected with
 * PFF_ERR_INVALID and a message.  Allocates nothing.  The first call on each
 * device looks up the array's device address (with that device current) and
 * should come before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (different streams, no ordering) race; the leftover
 * contents of earlier calls are never read. */
int pff_chebyshev_smooth_noalloc(pff_level* level, pff_prec prec, int degree, double lmin, double lmax,
                                 const void* diag, const void* b, void* x, void* stream);

/* ----------------------------------------------------------------------------
 * Newton-Krylov solver with p-multigrid preconditioning (Sec. 5: Newton, GMRES
 * with adaptive classical Gram-Schmidt refinement, p-multigrid with Chebyshev
 * smoothing; the paper's AMG coarse solve is replaced by GMRES on the assembled
 * order-1 Galerkin operator, preconditioned by a geometric h-multigrid V-cycle
 * on its structured grid (coarse_solver 2, the default; Jacobi-preconditioned
 * GMRES and Chebyshev-Jacobi remain as 1 and 0)).  Outer iterations, Krylov vectors and
 * inner products are FP64; with mixed = 1 the level operators and smoothers run
 * in FP32 (stored tangent copied by pff_op_enable_f32), and the assembled
 * coarsest level is built and applied in FP32 arithmetic (element matrices from
 * the FP32 words, FP32 copy of the stencil for its products; FP64 storage, FP64
 * vectors and FP64 GMRES); the adjoint's transposed coarse products stay FP64.
 * ------------------------------------------------------------------------- */
typedef struct pff_solver pff_solver;

typedef struct {
  int mixed;            /* 1: FP32 multigrid levels and smoothers; 0: all FP64 */
  int cheb_degree;      /* Chebyshev degree of pre- and post-smoothing */
  double cheb_lo;       /* smoothing interval [cheb_lo, cheb_hi] * lambda_max(D^-1 J) */
  double cheb_hi;
  int coarse_degree;    /* Chebyshev degree of the coarsest-level solve */
  double coarse_lo;     /* coarse interval [coarse_lo, cheb_hi] * lambda_max */
  int power_iters;      /* Arnoldi steps estimating lambda_max(D^-1 J) per level (<= restart) */
  int krylov_restart;   /* FGMRES restart length, 1..60 */
  int krylov_maxit;     /* iterations per linear solve */
  double krylov_rtol;   /* relative tolerance of each linear solve */
  int newton_maxit;     /* Newton iterations per call */
  double newton_rtol;   /* stop when ||r|| <= newton_rtol * ||r_0|| */
  int line_search_max;  /* step halvings of the backtracking line search (0 = full steps) */
  int coarse_solver;    /* coarsest assembled level: 0 Chebyshev(coarse_degree), 1 Jacobi-GMRES,
                           2 GMRES preconditioned by a geometric h-multigrid V-cycle (full
                           coarsening of the Q1 grid while the element counts are even and
                           >= 4; Galerkin element matrices, trilinear transfers,
                           Chebyshev(cheb_degree) smoothing, Chebyshev(coarse_degree) on
                           the coarsest grid) */
  double coarse_rtol;   /* coarse GMRES relative tolerance */
  int coarse_maxit;     /* coarse GMRES iterations per coarse solve */
  int verbose;          /* 1: one line per Newton iteration on stderr */
  int outer_prec;       /* fine-level action inside FGMRES: PFF_F64, or PFF_DF64 (pff_op_enable_df) */
  int newton_stall;     /* give up (converged = 0) once ||r|| fell by less than 2x over this many
                           Newton iterations, so that a load-step cut-back starts early; 0 = never */
  int eig_every;        /* re-estimate the lambda_max bounds every eig_every-th Newton iteration of a
                           solve (1 = every one); 0 = only on the first (later ones reuse them) */
  int level_words;      /* mixed = 1: stored words of the FP32 level actions and smoothers, 32 (the FP32
                           copy) or 16 (BF16 words, PFF_F32_BF16; needs pff_op_enable_bf16) */
} pff_solver_params;

typedef struct {
  int newton_iterations;
  int krylov_iterations;    /* summed over the Newton iterations */
  int converged;
  int status;               /* kernel status bits of a failed residual */
  int line_search_cuts;     /* step halvings taken by the line search */
  int coarse_iterations;    /* coarsest-level Krylov iterations, summed */
  double res0, res;         /* ||r|| at the first and the last residual */
  double last_krylov_relres;
  double t_residual, t_setup, t_krylov;  /* seconds, host clock around synchronised phases */
  double res_history[64];   /* ||r|| per Newton iteration */
} pff_newton_stats;

/* Fills the defaults: mixed 1, Chebyshev(3) on [0.1, 1.1] lambda_max, coarsest
 * assembled level solved by GMRES to 1e-2 (at most 200 iterations)
 * preconditioned by one h-multigrid V-cycle (coarse_solver 2; Chebyshev(16)
 * on [0.02, 1.1] on its coarsest grid), 10 Arnoldi steps,
 * FGMRES(30) to 1e-3 with at most 200 iterations, Newton to 1e-8 in at most 20
 * iterations with up to 8 line-search halvings, quiet. */
int pff_solver_default_params(pff_solver_params* params);
/* levels[0] = the fine level of op (pff_create_level with the fine order), then
 * coarser levels with decreasing order; if the last has order 1 its operator is
 * assembled (27-point stencil, 4x4 blocks, FP64).  Allocates the level vectors,
 * the FGMRES basis ((restart + 1) + restart fine vectors) and work space. */
int pff_create_solver(pff_op* op, int nlevels, pff_level* const* levels, const pff_solver_params* params,
                      pff_solver** solver);
int pff_destroy_solver(pff_solver* solver);
/* Diagonals, coarse assembly and lambda_max estimates for the current stored
 * linearisation (call after pff_residual).  Synchronises the stream. */
int pff_solver_setup(pff_solver* solver, void* stream);
/* lambda_max of D^-1 J estimated for a level by the last setup (spectral radius of
 * the Hessenberg matrix of power_iters Arnoldi steps from a seeded random-sign
 * vector; power iteration on the assembled coarsest level). */
int pff_solver_level_lambda(const pff_solver* solver, int level, double* lmax);
/* One V-cycle z = M^-1 r on FP64 fine vectors. */
int pff_solver_vcycle(pff_solver* solver, const double* r, double* z, void* stream);
/* y = A_c x with the assembled coarse operator (FP64 coarse vectors). */
int pff_solver_coarse_apply(pff_solver* solver, const double* x, double* y, void* stream);
/* Geometric h-hierarchy of coarse_solver 2 (level 0 = the assembled Q1 level;
 * valid after pff_solver_setup): number of levels (0 without the hierarchy). */
int pff_solver_num_hlevels(const pff_solver* solver);
/* Element grid (dims[3], host) and lambda_max(D^-1 A_l) estimate of h-level l. */
int pff_solver_hlevel_info(const pff_solver* solver, int level, int* dims, double* lmax);
/* y = A_l x on h-level l (FP64 [4][N_n(l)] device vectors): the Galerkin
 * operator P^T A_(l-1) P with the Dirichlet DoFs of the level set to identity. */
int pff_solver_hlevel_apply(pff_solver* solver, int level, const double* x, double* y, void* stream);
/* One h-multigrid V-cycle x = M_h^-1 b on h-level 0 (FP64 Q1-level vectors). */
int pff_solver_hcycle(pff_solver* solver, const double* b, double* x, void* stream);
/* FGMRES solve J x = b (x starts at 0); returns iterations and ||b - J x|| / ||b||. */
int pff_solver_krylov(pff_solver* solver, const double* b, double* x, double rtol, int maxit, int* iters,
                      double* relres, void* stream);
/* Newton iterations on z (FP64 [4][N_n], Dirichlet values already imposed):
 * residual, setup, FGMRES to krylov_rtol, backtracking line search on z - alpha dz
 * (a residual with det F <= 0 or non-finite values counts as a rejected step),
 * until newton_rtol.  The last residual evaluated is at the returned z. */
int pff_newton_solve(pff_solver* solver, double* z, pff_newton_stats* stats, void* stream);

/* One reverse step of the discrete adjoint of a load-step sequence (the paper
 * derives no adjoint; this extends its linearisation, App. B/C, to the
 * committed history and the phase parameters).  For step n with converged
 * state z_n (device FP64 [4][N_n]) and committed history of the previous step
 * hist_prev (device [15][N_q]), reaction F_n = sum of the internal force over
 * the DoFs selected by sel (device uint8 [4][N_n]) and dL/dF_n = wF:
 *   recompute the linearisation at (z_n, hist_prev) (the operator's committed
 *   history becomes hist_prev), solve J_n^T lam = wF J_int^T sel +
 *   (dPhi/dz)^T hbar_n (Dirichlet entries zero) by FGMRES to rtol with the
 *   transposed p-multigrid cycle, then
 *   hbar_prev = (wF sel - lam)^T dR/dh + hbar_n^T dPhi/dh   (device [15][N_q]) and
 *   grad[6 k + j] += (wF sel - lam)^T dR/dtheta_kj + hbar_n^T dPhi/dtheta_kj
 * with theta_k = (E_inf, nu_inf, sigma0, eta_d, Gc, l0) of phase k (grad: HOST
 * array of 6 nphase doubles).  hbar_n = NULL means zero (last step).  Phi is the
 * trial history map, R the residual.  Synchronises the stream. */
int pff_adjoint_step(pff_solver* solver, const double* z, const double* hist_prev, const uint8_t* sel, double wF,
                     const double* hbar_n, double* hbar_prev, double* grad, double rtol, int maxit, int* iters,
                     void* stream);

/* y = a x + b y on n entries of the given precision (device vectors). */
int pff_vec_axpby(pff_prec prec, int64_t n, double a, const void* x, double b, void* y, void* stream);

/* Accept the trial history written by the last pff_residual (Box 1 step 4,
 * C_in^-1 = F^-1 exp(2 eps_e) F^-T; eps_p += dgamma; H = max(H_n, psi+);
 * phi_n = phi). */
int pff_commit_history(pff_op* op, void* stream);
/* Copies of the per-point data (device destinations). which = 0 committed, 1 trial. */
int pff_get_history(pff_op* op, int which, double* hist, void* stream);
/* Per-point decision flags of the last pff_residual (uint8 [N_q], device
 * destination): bit 0 the Prandtl branch yielded (Box 1 step 2), bit 1 the
 * crack-driving history was raised (psi+ > H_n), bit 2 the tensile branch of
 * the energy split (theta >= 0). */
int pff_get_flags(pff_op* op, uint8_t* flags, void* stream);
/* Copy of the stored linearisation in the canonical point order: out[67][N_q]
 * (device FP64); for tests and diagnostics. */
int pff_get_linearization(pff_op* op, double* out, void* stream);

/* Synchronises `stream`, returns the kernel status bits accumulated since the
 * last call in *status and clears them. */
int pff_get_status(pff_op* op, void* stream, int* status);
/* Summary of the state for a load-step log (Sec. 5 reports reaction curves,
 * plastic strain and damage fields): out8 (HOST, 8 doubles) = numbers of
 * quadrature points whose flags of the last residual have the yield, history
 * active and theta >= 0 bits; largest and smallest nodal phase field of z
 * (device FP64 [4][N_n]); nodes with phi > 0.9; largest accumulated plastic
 * strain and largest history field H of the committed history.  Synchronises
 * the stream. */
int pff_state_summary(pff_op* op, const double* z, double* out8, void* stream);

/* Pipe-rate probe (measurement aid; the paper has no counterpart): launches
 * `blocks` x `threads` threads that each run 8 independent dependent chains of
 * `iters` multiply-adds on one arithmetic pipe, and returns in *flops the
 * floating-point operations that launch performs, so that flops / (launch
 * time) is the pipe's throughput on this GPU at its current clocks:
 *   PFF_PROBE_DFMA  FP64 FMA (2 flop each), PFF_PROBE_FFMA  FP32 FMA,
 *   PFF_PROBE_DMMA  FP64 tensor-core mma.sync m8n8k4 (512 flop per warp op),
 *   PFF_PROBE_CVT   FP64 -> FP32 -> FP64 conversion instructions (*flops then
 *                   counts conversions, two per chain step).
 * sink: device FP64 [blocks * threads] receiving the chains' final sums
 * (keeps them live).  Asynchronous on the stream; iters a multiple of 4,
 * threads a multiple of 32 in [32, 1024]; PFF_ERR_INVALID otherwise. */
#define PFF_PROBE_DFMA 0
#define PFF_PROBE_FFMA 1
#define PFF_PROBE_DMMA 2
#define PFF_PROBE_CVT 3
int pff_probe_pipe(int kind, int64_t iters, int blocks, int threads, double* sink, double* flops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PFF_H */
