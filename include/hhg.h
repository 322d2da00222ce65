/*
 * hhg.h -- C ABI of libhhgs: scaled-stencil P1 finite element operators for
 * vector-valued PDEs on hierarchical hybrid grids, on one sm_103a GPU.
 *
 * The method is the "physical stencil scaling" of Drzisga, Ruede and Wohlmuth,
 * "Stencil scaling for vector-valued PDEs on hybrid grids with applications to
 * generalized Newtonian fluids" (arXiv 1908.08666):
 *   - the domain is an unstructured mesh of macro tetrahedra, each refined
 *     uniformly (Sec. 2, Bey's rule);
 *   - inside a macro every node sees the same 15-point stencil of 3x3 blocks
 *     (Sec. 2.4, Fig. subtypes_and_stencil);
 *   - for a nodal coefficient k the off-centre block of the edge (i, j) is
 *       S_ij = khat_ij * Shat_ij + R_ij                     (Lemma 2.1)
 *     with the patch mean khat (eq. patchmean) and the antisymmetric
 *     correction R_ij = sum_c (k_{r_c} - k_{r_c^m}) S^c_ij (eq. correctionterm3D);
 *     the centre block is minus the row sum;
 *   - rows of nodes on macro faces/edges/vertices follow the interface
 *     definition of Sec. 2.2.
 *
 * Conventions used by every entry point below.
 *
 * Layout.  A level stores each macro's closed tetrahedral lattice
 * {(i,j,k): i,j,k >= 0, i+j+k <= n}, n = 2^level, in compact order
 *     idx(i,j,k) = S(k) + R_k(j) + i,   S(k) = T(n+1) - T(n+1-k),
 *     R_k(j) = j (2(n-k) + 3 - j) / 2,  T(a) = a(a+1)(a+2)/6,
 * macros concatenated (macro m starts at m * T(n+1)); hhg_num_nodes returns
 * the number of entries E = M * T(n+1).  Lattice point (i,j,k) of macro m
 * with vertices (v0,v1,v2,v3) sits at v0 + (i(v1-v0) + j(v2-v0) + k(v3-v0))/n.
 * A vector field is stored component-major: component c of entry e at
 * [c*E + e] (3 components for velocity/displacement).  A scalar field
 * (coefficient, pressure) has one component.  Nodes on the macro skeleton
 * appear once per incident macro; every routine that writes a field writes
 * all copies identically, and every input field must have consistent copies
 * (hhg_scatter_unique produces such fields).
 *
 * Pointers.  Arguments named *_dev are device pointers owned by the caller,
 * sized as stated; *_host are host pointers.  The library owns everything
 * else (mesh, stencils, hierarchy, workspaces) and frees it in hhg_destroy.
 *
 * Execution.  All device work runs on the stream given to hhg_create, in
 * order.  Calls that return host scalars wait for the stream with a bounded
 * wait (hhg_set_timeout) and return HHG_ERR_TIMEOUT when it runs out.
 *
 * Errors.  Every call returns an hhg_status; nothing aborts.  hhg_last_error
 * gives a message for the last failing call on the context.
 *
 * Dirichlet rows.  x holds the Dirichlet values at Dirichlet nodes.  The
 * operator applied to x returns x on Dirichlet rows (identity rows, columns
 * kept); residuals are 0 there.
 */
#ifndef HHG_H
#define HHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hhg_ctx hhg_ctx;

typedef enum {
  HHG_OK = 0,
  HHG_ERR_ARG = 1,
  HHG_ERR_CUDA = 2,
  HHG_ERR_OOM = 3,
  HHG_ERR_UNSUPPORTED = 4,
  HHG_ERR_NOT_CONVERGED = 5,
  HHG_ERR_NUMERIC = 6,
  HHG_ERR_TIMEOUT = 7,
  HHG_ERR_STATE = 8
} hhg_status;

/* Arithmetic type of a call's vectors. */
typedef enum { HHG_F64 = 0, HHG_F32 = 1, HHG_BF16 = 2 } hhg_dtype;

/* Operator families (Sec. 5.1.2 elasticity, Sec. 5.2 Stokes). */
typedef enum { HHG_ELASTICITY = 0, HHG_STOKES = 1 } hhg_problem_kind;

/* Sec. 2: physical scaling (Lemma 2.1), unphysical scaling (eq.
 * stencilscalingwithoutcorr, R = 0), or nodal integration everywhere
 * (eq. nodalintegration; elasticity only): the paper's comparison method, whose
 * macro-interior rows sum kbar^t times the element stiffness over the 24 elements
 * around each node on the fly (skeleton rows are a_h rows in every variant's
 * practical interface rule; hhg_residual_noalloc rejects this variant).
 * STORED (elasticity only) is the physical-scaling operator with the macro-interior rows
 * stored, the paper's third method of Sec. 4 (Table memorytotal: 135 values per node):
 * the first sweep on a level and precision after hhg_set_problem or hhg_set_coefficient
 * computes the 15 3x3 blocks of every macro-interior row (in FP64 from the FP64
 * coefficient, rounded to the sweep's precision; 135 * E values of that precision per
 * level, owned by the library) and later sweeps read them; skeleton rows are computed
 * as for PHYSICAL.  The operator equals PHYSICAL's up to rounding. */
typedef enum { HHG_PHYSICAL = 0, HHG_UNPHYSICAL = 1, HHG_NODAL = 2, HHG_STORED = 3 } hhg_variant;

/* khat: patch mean (eq. patchmean) or edge mean (k_i + k_j)/2 (Remark after Sec. 2.2). */
typedef enum { HHG_KHAT_PATCH = 0, HHG_KHAT_EDGE = 1 } hhg_khat;

/* Sec. 2.2 interface rows: SYMMETRIC uses a_h for pairs of skeleton nodes and
 * the scaled block otherwise, with a zero-row-sum centre block on skeleton
 * rows; PRACTICAL uses the a_h row for every skeleton node. */
typedef enum { HHG_IFACE_SYMMETRIC = 0, HHG_IFACE_PRACTICAL = 1 } hhg_iface;

typedef struct {
  hhg_problem_kind kind;
  double nu;          /* Poisson ratio (elasticity): a^{E=1} = 1/(1+nu)(eps,eps) + nu/((1+nu)(1-2nu))(div,div) */
  hhg_variant variant;
  hhg_khat khat;
  hhg_iface iface;
} hhg_problem;

/* Create a context on CUDA device `device`; all work is issued on `cuda_stream`
 * (a cudaStream_t, may be NULL for the legacy default stream). */
hhg_status hhg_create(hhg_ctx** ctx, int device, void* cuda_stream);
hhg_status hhg_destroy(hhg_ctx* ctx);
const char* hhg_last_error(hhg_ctx* ctx);
/* Bound for every host wait on the stream, in milliseconds (default 120000). */
hhg_status hhg_set_timeout(hhg_ctx* ctx, int64_t milliseconds);

/* Macro mesh T_H (Sec. 2): nverts vertices xyz_host[3*nverts], ntets tetrahedra
 * tets_host[4*ntets] (vertex ids; the order of each tetrahedron's vertices fixes
 * its refinement, Bey's rule).  dirichlet_face_flags_host is NULL (every face of
 * exactly one macro is Dirichlet) or int32[4*ntets]: face f of tetrahedron t
 * (the face opposite its vertex f) is Dirichlet when non-zero.  Errors: ARG for
 * degenerate tetrahedra or bad ids. */
hhg_status hhg_set_macro_mesh(hhg_ctx* ctx, const double* xyz_host, int64_t nverts, const int64_t* tets_host,
                              int64_t ntets, const int32_t* dirichlet_face_flags_host);

/* Build levels coarsest..level_max (n = 2^level intervals per macro edge; the
 * coarsest level is 2 unless hhg_set_coarsest_level chose another; level 2 has
 * one interior node per macro).  Errors: ARG unless coarsest <= level_max <= 9. */
hhg_status hhg_refine(hhg_ctx* ctx, int level_max);

/* Coarsest level of the hierarchy that hhg_refine builds, and so of every
 * multigrid cycle (Sec. 5: the coarsest grid is solved directly): 0 (the macro
 * mesh itself), 1 (plus the edge midpoints: no macro-interior or face-interior
 * nodes) or any level up to 9; default 2.  Meshes of many macros need 0 or 1,
 * since the direct coarse solve takes at most 3000 free DoFs (elasticity: 3 per
 * free node; Stokes: 3 per free node plus one pressure per node).  Call it after
 * hhg_set_macro_mesh (which resets it to 2) and before hhg_refine.  Errors: ARG
 * outside [0, 9]; STATE when the levels are already built. */
hhg_status hhg_set_coarsest_level(hhg_ctx* ctx, int level);

/* Select the operator (computes the per-macro reference stencils Shat and the
 * correction stencils S^1..3 of eq. correctionterm3D from element stiffness
 * in FP64 on the host, and uploads them). */
hhg_status hhg_set_problem(hhg_ctx* ctx, const hhg_problem* problem);

/* Sizes of a level: entries (vector length E), unique nodes, free (non-Dirichlet) nodes. */
hhg_status hhg_num_nodes(hhg_ctx* ctx, int level, int64_t* entries, int64_t* unique_nodes, int64_t* free_nodes);

/* Coordinates of every entry of a level: xyz_host[3*E] (row per entry). */
hhg_status hhg_entry_coords(hhg_ctx* ctx, int level, double* xyz_host);
/* Unique node of every entry: map_host[E]; unique nodes are numbered macro
 * interiors first (macro by macro, compact order), then skeleton nodes.
 * dirichlet_host (nullable) receives int8[unique] Dirichlet flags. */
hhg_status hhg_entry_to_unique(hhg_ctx* ctx, int level, int64_t* map_host, int8_t* dirichlet_host);

/* Field conversion between the library layout and unique-node order.
 * gather: dst_dev[c*U + u] = src_dev[c*E + first entry of u]; scatter: the
 * reverse, writing every copy.  comps = 1 or 3 (or 4 for Stokes velocity+pressure
 * stored as 4 components). */
hhg_status hhg_gather_unique(hhg_ctx* ctx, int level, hhg_dtype dt, int comps, const void* src_dev, void* dst_dev);
hhg_status hhg_scatter_unique(hhg_ctx* ctx, int level, hhg_dtype dt, int comps, const void* src_dev, void* dst_dev);

/* Nodal coefficient k (E for elasticity, mu for Stokes; Sec. 2, eq. nodalquad)
 * on the finest level, k_dev[E] in the library layout (dtype F64, F32 or BF16; BF16
 * values are IEEE bfloat16 bit patterns, uint16).  Coarser levels receive the
 * injection (coarse nodes are fine nodes).  With BF16 the operator is the one of the
 * BF16 coefficient on every path; FP32 sweeps then read the coefficient of macro-interior
 * nodes as BF16 (2 instead of 4 bytes per node), the other kernels read the same values
 * widened.  The error against the FP32/FP64 coefficient is that of rounding each nodal
 * k to BF16 (relative error at most 2^-8): each scaled block changes by at most 2^-8
 * times the sum of the magnitudes of its terms. */
hhg_status hhg_set_coefficient(hhg_ctx* ctx, const void* k_dev, hhg_dtype dt);

/* y = A x on `level` (eq. residuallinalg without f): x_dev, y_dev are 3*E
 * vectors of type dt; Dirichlet rows return x. */
hhg_status hhg_apply(hhg_ctx* ctx, int level, hhg_dtype dt, const void* x_dev, void* y_dev);

/* r = f - A x on free rows, 0 on Dirichlet rows (eq. residuallinalg).
 * norm2_host (nullable) receives sum over unique free nodes of |r|^2 in FP64
 * (this waits for the stream). */
hhg_status hhg_residual(hhg_ctx* ctx, int level, hhg_dtype dt, const void* f_dev, const void* x_dev, void* r_dev,
                        double* norm2_host);

/* ---------------------------------------------------------------------------
 * Smoothers, multigrid and solvers.  Sec. 5 solves with geometric multigrid:
 * linear interpolation and its transpose between levels, coarse operators by
 * rediscretisation with the injected coefficient, a smoother on every level
 * and a coarse-grid solve; this library uses point-Jacobi or Chebyshev
 * smoothing (bounds [lo, hi] * lambda_max(D^-1 A), lambda_max from power
 * iterations) and an exact dense solve on the coarsest level (level 2).
 * ------------------------------------------------------------------------- */
/* HYBRID_GS is the paper's smoother (Sec. 5): Gauss-Seidel inside the macros, Jacobi-like
 * across their interfaces.  One step: a point-Jacobi step with weight omega on every node of
 * the macro skeleton (faces, edges, vertices of the macro mesh), then Gauss-Seidel over the
 * macro-interior nodes in eight colour passes, colour 4 (i % 2) + 2 (j % 2) + (k % 2) of the
 * node's lattice coordinates in its macro, in that order, each node taking the newest values
 * (no two nodes of a colour are neighbours, so a pass updates them all at once). */
typedef enum { HHG_SMOOTH_JACOBI = 0, HHG_SMOOTH_CHEBYSHEV = 1, HHG_SMOOTH_HYBRID_GS = 2 } hhg_smoother;
/* Coarse-level coefficient: injection (the reading of Sec. 5's rediscretisation),
 * or a local arithmetic / harmonic mean of the finer level's (for large jumps). */
typedef enum { HHG_COARSE_INJECT = 0, HHG_COARSE_MEAN = 1, HHG_COARSE_HARMONIC = 2 } hhg_coarse_coeff;

typedef struct {
  hhg_smoother smoother;
  int pre, post;          /* smoothing steps before / after the coarse correction (default 2, 2) */
  double omega;           /* Jacobi damping (also of the skeleton step of HYBRID_GS) */
  double cheby_lo, cheby_hi; /* Chebyshev interval as fractions of lambda_max (default 1/8, 1.1) */
  int power_iters;        /* power iterations for lambda_max */
  hhg_coarse_coeff coarse_coeff; /* coefficient of the coarse levels (default injection) */
  /* Stokes inexact-Uzawa multigrid (HHG_SOLVE_STOKES_UZAWA*): V(uzawa_pre, uzawa_post)
   * with uzawa_extra more steps on every coarser level (variable V-cycle, default 3, 3, 2);
   * each Uzawa step smooths the velocity with uzawa_vsteps steps of the smoother above
   * (default 2) and then relaxes the pressure with weight uzawa_omega (default 0.5). */
  int uzawa_pre, uzawa_post, uzawa_extra, uzawa_vsteps;
  double uzawa_omega;
} hhg_mg_params;

hhg_status hhg_set_mg_params(hhg_ctx* ctx, const hhg_mg_params* params);
/* Diagonals, lambda_max of every level (unless set) and the dense coarse inverse
 * (at most 3000 coarse DoFs).  With coarse_coeff = MEAN or HARMONIC it first replaces
 * the coarse levels' coefficient (level by level from the finest): at a coarse
 * macro-interior node, the weighted mean of the fine coefficient (or of its inverse)
 * over the node and its 14 fine neighbours with weights 1 and 1/2 (the restriction's
 * weights, normalised); skeleton nodes keep the injected value.  Call after
 * hhg_set_coefficient; waits for the stream. */
hhg_status hhg_mg_setup(hhg_ctx* ctx);
hhg_status hhg_get_lambda_max(hhg_ctx* ctx, int level, double* lambda);
hhg_status hhg_set_lambda_max(hhg_ctx* ctx, int level, double lambda);
/* Point diagonal of A on `level` (3*E, 1 on Dirichlet rows). */
hhg_status hhg_diagonal(hhg_ctx* ctx, int level, hhg_dtype dt, void* d_dev);
/* `steps` smoothing steps for A x = f on `level`, x updated in place (3*E). */
hhg_status hhg_smooth(hhg_ctx* ctx, int level, hhg_dtype dt, int steps, const void* f_dev, void* x_dev);
/* xf += P xc (linear interpolation from fine_level-1 to fine_level). */
hhg_status hhg_prolongate_add(hhg_ctx* ctx, int fine_level, hhg_dtype dt, const void* xc_dev, void* xf_dev);
/* rc = P^T rf (rc on fine_level-1; 0 on Dirichlet nodes). */
hhg_status hhg_restrict(hhg_ctx* ctx, int fine_level, hhg_dtype dt, const void* rf_dev, void* rc_dev);
/* One V(pre, post) cycle for A x = f on `level`, x updated in place. */
hhg_status hhg_vcycle(hhg_ctx* ctx, int level, hhg_dtype dt, const void* f_dev, void* x_dev);

typedef enum {
  HHG_SOLVE_PCG_JACOBI = 0, /* point-Jacobi preconditioned CG */
  HHG_SOLVE_MG_CG = 1,      /* CG preconditioned by one V-cycle */
  HHG_SOLVE_IR_MG_CG = 2,   /* FP64 iterative refinement around FP32 MG-CG (f, x in FP64) */
  HHG_SOLVE_MG = 3,         /* stationary V-cycles */
  /* Stokes (problem kind HHG_STOKES; f, x hold (u, v, w, p), 4*E values): MINRES
   * preconditioned by blockdiag(one velocity V-cycle, S^-1) with the diagonal Schur
   * surrogate S_ii = m_i / mu_i + (-C)_ii (m the lumped pressure mass, C the pressure
   * stabilisation); the pressure is shifted to zero mean (sum m_i p_i = 0) at the end. */
  HHG_SOLVE_STOKES_MINRES = 4,
  HHG_SOLVE_STOKES_IR_MINRES = 5, /* FP64 iterative refinement around FP32 MINRES */
  /* Elasticity on a mesh whose nodes lie on an axis-aligned uniform lattice: FP64
   * iterative refinement around FP32 flexible CG preconditioned by one V-cycle plus the
   * learned correction (hhg_learn_*; parameters must be set), or by the V-cycle alone
   * (IR_FCG, the same solver without the network). */
  HHG_SOLVE_IR_FCG_LEARNED = 6,
  HHG_SOLVE_IR_FCG = 7,
  /* Stokes: the inexact Uzawa multigrid of Sec. 5.2 -- all-at-once V-cycles on the saddle
   * system (velocity and pressure restricted and prolongated together, coarsest level
   * solved exactly), each smoothing step a velocity smoothing with the pressure fixed
   * followed by the pressure update p -= omega S^-1 (g - B u - C p) with S as for MINRES.  UZAWA
   * iterates V-cycles in the type of f and x; IR_UZAWA refines in FP64 around FP32
   * V-cycles, each inner solve to inner_rtol (at most inner_max_iter cycles).  The
   * pressure is shifted to zero mean at the end. */
  HHG_SOLVE_STOKES_UZAWA = 8,
  HHG_SOLVE_STOKES_IR_UZAWA = 9,
  /* Stokes on a mesh whose nodes lie on an axis-aligned uniform lattice: FP64 iterative
   * refinement around FP32 flexible GCR (generalised conjugate residual with a variable
   * preconditioner: each new direction is made K^T K-orthogonal to the stored ones and the
   * step minimises |r|_2; equal to flexible GMRES in exact arithmetic; restarted after 30
   * directions), preconditioned by one inexact Uzawa V-cycle from zero (as
   * HHG_SOLVE_STOKES_UZAWA) plus the learned correction (hhg_learn_*; parameters must be
   * set), or by the V-cycle alone (IR_FGCR).  Each inner solve runs to inner_rtol (at most
   * inner_max_iter applications); the pressure is shifted to zero mean at the end. */
  HHG_SOLVE_STOKES_IR_FGCR_LEARNED = 10,
  HHG_SOLVE_STOKES_IR_FGCR = 11
} hhg_solve_method;

typedef struct {
  hhg_solve_method method;
  int level;
  hhg_dtype dt;        /* type of f and x (F64 required for IR_MG_CG) */
  double rtol;         /* stop when |f - A x| <= rtol |f - A x0| (2-norm over free unique DoFs) */
  int max_iter;
  double inner_rtol;   /* IR: relative tolerance of each FP32 inner solve */
  int inner_max_iter;
} hhg_solve_opts;

typedef struct {
  int iterations;        /* outer iterations (CG / V-cycles / refinement steps) */
  int inner_iterations;  /* IR: total inner CG iterations */
  double residual0;      /* |f - A x0| */
  double rel_residual;   /* final |f - A x| / |f - A x0|, in the type of x */
  double seconds;        /* host wall time of the call */
  int converged;
} hhg_solve_report;

/* Solve A x = f on opts->level (x holds the initial guess and the Dirichlet
 * values).  Returns HHG_ERR_NOT_CONVERGED (with x and the report filled) when
 * max_iter is reached, HHG_ERR_NUMERIC on a non-finite residual. */
hhg_status hhg_solve(hhg_ctx* ctx, const hhg_solve_opts* opts, const void* f_dev, void* x_dev,
                     hhg_solve_report* report);

/* Stokes saddle operator (problem kind HHG_STOKES, Sec. 5.2): on (u, v, w, p)
 * vectors of 4*E values (component-major),
 *     K = [[A(mu), B^T], [B, C]],  A(mu) = scaled-stencil operator of (2 mu eps(u), eps(v)),
 *     B = -(div u, q),  C = -(h^2/12) (grad p, grad q),  h = (6 |T|)^{1/3} / n per macro,
 * mu = the coefficient.  Velocity-Dirichlet rows are identity rows (residual 0);
 * every pressure row is free. */
hhg_status hhg_stokes_apply(hhg_ctx* ctx, int level, hhg_dtype dt, const void* x_dev, void* y_dev);
hhg_status hhg_stokes_residual(hhg_ctx* ctx, int level, hhg_dtype dt, const void* f_dev, const void* x_dev,
                               void* r_dev, double* norm2_host);

/* ---------------------------------------------------------------------------
 * Generalised Newtonian (Carreau) Stokes, Sec. 5.2.2 and Sec. 3.
 * ------------------------------------------------------------------------- */
typedef struct {
  double eta0, eta_inf, kappa, r; /* mu = eta_inf + (eta0 - eta_inf) (1 + kappa |eps(u)|^2)^r (eq. carreau) */
} hhg_carreau;

/* Nodal viscosity from a velocity field (Sec. 3): at every node the affine
 * least-squares fit of each velocity component over the node and its mesh
 * neighbours (eq. minimization_problem, m = 1; on macro interiors the patch is
 * point-symmetric and the fit reduces to a fixed slope operator) gives grad u,
 * |eps(u)|^2 = eps : eps, and mu by the Carreau law.  u_dev: FP64, components
 * at u_dev[c*E + e] (c = 0..2; a Stokes vector can be passed directly);
 * mu_dev: FP64[E], every copy written. */
hhg_status hhg_carreau_viscosity(hhg_ctx* ctx, int level, const hhg_carreau* params, const void* u_dev,
                                 void* mu_dev);

/* Boundary traction (Neumann) load, the term int_{Gamma_N} t . v ds of the weak form
 * (Sec. 5.1.3, the traction on the foam block's top plane): f += M_Gamma t on the free
 * rows, with M_Gamma the exact P1 mass matrix of the refined triangles of the flagged
 * macro faces and t the nodal traction interpolated on them.  face_flags_host: int32[4 *
 * ntets], face f of tetrahedron t (the face opposite its vertex f) carries the traction
 * when non-zero; it must be a boundary face (ARG otherwise).  t_dev and f_dev: 3
 * components of stride E in dt (FP64 or FP32) at `level`; every copy of a node receives
 * the same value; Dirichlet rows are left unchanged.  Allocates temporaries and waits for
 * the stream. */
hhg_status hhg_traction_load(hhg_ctx* ctx, int level, hhg_dtype dt, const int32_t* face_flags_host,
                             const void* t_dev, void* f_dev);

/* 2D variant of the stencil scaling (Sec. 2.1, Sec. 2.3): y = A x for the vector P1
 * operator of E (1/(1+nu) (eps(u), eps(v)) + nu/((1+nu)(1-2nu)) (div u, div v)) on one
 * macro triangle tri_host[6] = (x0, y0, x1, y1, x2, y2) refined uniformly to n = 2^level
 * intervals per edge (level 1..14), with the scaled 7-point stencil of 2x2 blocks: per
 * interior edge khat Shat plus, for variant HHG_PHYSICAL, the correction of eq.
 * corrtermgeneral, whose antisymmetric block does not depend on the triangle's shape (eq.
 * correction2d); HHG_UNPHYSICAL drops it; HHG_NODAL applies nodal integration a_h (each
 * element block scaled by its element's vertex mean), the comparison method.  Lattice points (i, j), i + j <= n, at v0 + (i (v1 -
 * v0) + j (v2 - v0)) / n, index j (n + 1) - j (j - 1) / 2 + i, N = (n+1)(n+2)/2 of them;
 * k_dev[N] the nodal coefficient, x_dev and y_dev 2 components of stride N (component-
 * major), all in dt (FP64 or FP32) on the device.  The triangle's boundary is Dirichlet
 * (y = x there).  Runs on the context's stream; needs no mesh.  Errors: ARG (null or
 * aliased pointers, level, nu, degenerate triangle, dtype), UNSUPPORTED (the STORED variant). */
hhg_status hhg_apply_2d(hhg_ctx* ctx, const double* tri_host, int level, double nu, int variant, hhg_dtype dt,
                        const void* k_dev, const void* x_dev, void* y_dev);

/* Degree m of the least-squares fit on the macro skeleton (eq. minimization_problem,
 * m in {1, 2}; default 1), used by hhg_carreau_viscosity and hhg_picard.  m = 2 fits a
 * quadratic in the monomials 1, x_a, x_a x_b over the node's patch where the patch
 * determines it (at least 10 points and every Cholesky pivot of the normal equations in
 * patch-scaled coordinates above 1e-10 of the largest diagonal entry) and the affine
 * polynomial elsewhere (one-sided patches on the domain boundary, where the quadratic
 * terms are not determined).  Macro-interior nodes keep the affine slope operator: on
 * their point-symmetric patches both fits have the same gradient (Sec. 3).  Errors: ARG
 * for another degree. */
hhg_status hhg_set_strain_fit(hhg_ctx* ctx, int degree);

typedef struct {
  hhg_carreau carreau;
  int level;
  double picard_tol;     /* stop when max_i |u_i - u_i_prev| < picard_tol * max_i |u_i| (Alg. 1) */
  int max_picard;
  double step_rtol;      /* relative tolerance of the inexact solve of each fixed-point step: one FP64
                            refinement step around FP32 MINRES to step_rtol; below 1e-6, FP64
                            refinement steps around FP32 MINRES to 1e-3 (at most 50) */
  int step_max_iter;     /* MINRES iterations per step */
  double final_rtol;     /* final solve to this relative residual (Alg. 1: 1e-3) */
} hhg_picard_opts;

typedef struct {
  int picard_iterations;
  int minres_iterations; /* total */
  double final_rel_residual;
  double last_change;    /* max |u - u_prev| / max |u| of the last fixed-point step */
  double mu_min, mu_max;
  double seconds;
  int converged;
} hhg_picard_report;

/* Alg. 1: fixed-point (Picard) iterations for Carreau Stokes on opts->level with FP64
 * f and x (4*E; x holds the initial guess and the Dirichlet velocity).  Each step sets
 * mu = mu(u) (FP64), refreshes the multigrid hierarchy, and solves the linearised saddle
 * system inexactly (FP64 refinement around FP32 MINRES); the final solve reaches
 * final_rtol and the viscosity is updated once more (left as the coefficient). */
hhg_status hhg_picard(hhg_ctx* ctx, const hhg_picard_opts* opts, const void* f_dev, void* x_dev,
                      hhg_picard_report* report);

/* Residual with norm that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * the time they need a residual norm -- a process whose device memory is owned
 * by another allocator (a caching allocator that has reserved the GPU, so a
 * cudaMalloc would fail), or a time-critical solver loop that must not pay
 * the latency and implicit device synchronisation of cudaMalloc/cudaFree.
 * It computes exactly what hhg_residual(ctx, level, dt, f_dev, x_dev, r_dev,
 * norm2_host) computes (r = f - A x on free rows, 0 on Dirichlet rows;
 * norm2_host = sum of |r|^2 over unique free nodes, FP64), with the caller's
 * inputs and outputs, but keeps its scratch (per-block partial sums and the
 * reduced value) in one static device array of 262,144 + 32 doubles (about
 * 2 MiB) that every GPU which loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine; the
 * context must already be set up (hhg_refine etc. allocate, this call does not).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process, so resetting the device (cudaDeviceReset) while the library is
 * loaded is not supported.  Every call waits for the stream (it polls the
 * stream with cudaStreamQuery after copying the norm to pinned host memory),
 * so it must not be called while the stream is being captured.  Levels whose residual needs more than 262,144 partial
 * sums (one per interior tile of each macro plus one per free skeleton node;
 * for the 6-macro cube: levels up to 7) are rejected with HHG_ERR_ARG.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other contexts on the same device) race on it.  The wait for the stream is
 * bounded (hhg_set_timeout). */
hhg_status hhg_residual_noalloc(hhg_ctx* ctx, int level, hhg_dtype dt, const void* f_dev, const void* x_dev,
                                void* r_dev, double* norm2_host);

/* ------------------------------------------------------------------------------------
 * Learned preconditioner.  Not part of the paper: a small convolutional network that
 * maps what a multigrid cycle leaves behind to a further correction, used inside flexible
 * CG (elasticity, nc = 3 unknowns per node) or flexible GCR (Stokes, nc = 4: velocity and
 * pressure).  Below, K is the system operator (A for elasticity, the saddle operator for
 * Stokes), MG(r) one V-cycle from zero for K e = r (the elasticity V-cycle, or the
 * inexact Uzawa V-cycle), and vectors have nc*E values.
 *
 * Grid.  The network runs on the node grid of a level: the mesh's nodes must lie on an
 * axis-aligned uniform lattice (Kuhn-split cubes, axis-aligned corner tetrahedra);
 * voxel (z, y, x) at index (z*H + y)*W + x holds that lattice point's node (empty voxels
 * are zero).  Other meshes get HHG_ERR_UNSUPPORTED.
 *
 * Network.  4 layers of 3x3x3 convolutions, 16 channels, zero padding, ReLU after the
 * first three; BF16 activations and weights, FP32 accumulation (tensor cores), FP32
 * biases and master weights.  hhg_learn_num_params() = 4*(27*16*16 + 16) parameters,
 * layer l at offset l*6928: W_l[t][i][o] at (t*16 + i)*16 + o (tap t = (dz+1)*9 +
 * (dy+1)*3 + (dx+1), input channel i, output channel o), then b_l[16].
 *
 * Input features per voxel (cin = 2 nc + 1 channels: 7 elasticity, 9 Stokes): r1/s (nc),
 * D z0/s (nc), log k - mean log k (1), where for a residual r: z0 = a0 v, v = MG(r),
 * with the energy-optimal step length a0 = (v, r)/(v, A v) for elasticity and a0 = 1 for
 * Stokes (the Uzawa cycle is a convergent iteration itself); r1 = r - K z0; D = point diagonal
 * of A (velocity) and, for the pressure, the diagonal Schur surrogate m_i/mu_i + (-C)_ii;
 * s = RMS of D z0 over the free DoFs (velocity at free nodes, pressure everywhere).
 * Output (nc channels): D c / s.  The preconditioned vector is z = a z0 + b c with
 * (a, b) minimising over span{z0, c} the energy norm of the error K^-1 r - z
 * (elasticity) or the residual norm |r - K z|_2 (Stokes), by 2x2 normal equations; when
 * that system is singular or not finite, z = z0.  An application never does worse in
 * that norm than the best multiple of the multigrid step alone.
 *
 * Training pairs.  From an error e: z0 as above for r = K e, e1 = e - z0 (Stokes: its
 * pressure shifted to zero mass-weighted mean), r1 = r - K z0; the pair is
 * (features(r1, z0), target D e1 / s).  hhg_learn_collect takes random errors (`cycles`
 * steps per e0, each continuing from e1); hhg_learn_collect_cg the errors of the plain
 * multigrid-preconditioned Krylov iterates.  Pairs take nc from the problem kind.
 * Loss: mean squared error over voxels and the nc output channels; Adam (0.9, 0.999,
 * 1e-8) with a cosine learning-rate decay to 5% of lr. */
int64_t hhg_learn_num_params(void);
/* Convolution kernel of the network: 0 = warp-level BF16 MMA (mma.sync m16n8k16) on a
 * shared-memory tile (default), 1 = 5th-generation tensor cores (tcgen05.mma with
 * accumulators in tensor memory, 6 x 27 MMAs of 128 x 16 x 16 per 32 x 4 x 4 output tile,
 * one tile per block), 2 = the same MMAs in a persistent pipeline (tensor-memory-
 * accelerator loads into two shared stages, two tensor-memory accumulator sets, an
 * epilogue warpgroup draining one while the next tile's MMAs run).  All give the same
 * results up to FP32 summation order. */
hhg_status hhg_learn_set_conv_kernel(hhg_ctx* ctx, int kernel);
/* Bound of the tensor-core convolution's (kernel 1) wait for its MMAs, in polls about 100 ns
 * apart; negative restores the default (2^24 polls).  Fault handling, not the paper: when the
 * wait runs out the kernel records an error, still waits (with the default bound) for the MMAs
 * it issued before freeing their tensor memory, skips its epilogue and returns; the call then
 * fails with HHG_ERR_TIMEOUT and the context falls back to convolution kernel 0.  A short
 * bound lets a test make the wait run out without a fault; the context stays usable. */
hhg_status hhg_learn_set_conv_wait(hhg_ctx* ctx, int64_t polls);
/* Coarse-grid mode (elasticity; levels = 0 default, 1..3): the network runs on the node
 * grid `levels` levels below the solve's.  Its inputs there are r1 restricted (P^T, as in
 * the V-cycle) and z0 injected (coarse nodes are fine nodes), D is that level's point
 * diagonal, and its correction is prolongated back (P, linear interpolation) before the
 * 2x2 combination; training pairs are stored on the coarse grid with the error injected
 * there.  Pairs keep the coarsening they were reserved with.  Errors: ARG for levels
 * outside 0..3, UNSUPPORTED for levels > 0 on a Stokes problem; an application, a pair
 * reservation or collection whose level minus the coarsening is below the coarsest level
 * fails with ARG, and collecting into pairs reserved with another coarsening with STATE. */
hhg_status hhg_learn_set_coarsening(hhg_ctx* ctx, int levels);
/* He-normal initialisation (std sqrt(2/(27*fan_in)), last layer x0.1; BF16 values,
 * zero biases) from a seeded generator, with the input and output channels of the
 * context's problem kind (7 / 3 elasticity, 9 / 4 Stokes); resets the optimiser state. */
hhg_status hhg_learn_init(hhg_ctx* ctx, uint64_t seed);
/* Copy the n = hhg_learn_num_params() FP32 parameters out of / into the context
 * (set: all must be finite; resets the optimiser state; weights are used in BF16). */
hhg_status hhg_learn_get_params(hhg_ctx* ctx, float* params_host, int64_t n);
hhg_status hhg_learn_set_params(hhg_ctx* ctx, const float* params_host, int64_t n);
/* Node-grid dimensions (D, H, W) of a level and its number of voxels with a free node. */
hhg_status hhg_learn_grid(hhg_ctx* ctx, int level, int* dhw_host, int64_t* free_voxels);
/* Input and output channels (cin, cout) of the context's problem kind (either pointer
 * nullable; no error beyond a null context). */
hhg_status hhg_learn_channels(hhg_ctx* ctx, int* cin_host, int* cout_host);
/* Network forward pass on B grids of D x H x W voxels: x_dev FP32 [B][D][H][W][cin]
 * (cin <= 16, rounded to BF16), out_dev FP32 [B][D][H][W][cout] (cout 3 or 4: the first
 * cout output channels). */
hhg_status hhg_learn_forward(hhg_ctx* ctx, const float* x_dev, int cin, int cout, int B, int D, int H, int W,
                             float* out_dev);
/* Loss against target_dev (FP32 [B][D][H][W][cout], cout 3 or 4) and its gradient with
 * respect to all parameters (grad_host: hhg_learn_num_params() floats, nullable), for
 * checking the backward pass.  Waits for the stream. */
hhg_status hhg_learn_loss_grad(hhg_ctx* ctx, const float* x_dev, int cin, const float* target_dev, int cout, int B,
                               int D, int H, int W, double* loss_host, float* grad_host);
/* Allocate storage for `capacity` training pairs of `level` (drops stored pairs). */
hhg_status hhg_learn_reserve_pairs(hhg_ctx* ctx, int level, int64_t capacity);
/* Append `cycles` pairs from the error e0_grid_dev (FP32 [D][H][W][nc] on the node grid
 * of `level`; velocity at Dirichlet nodes is ignored).  Needs hhg_mg_setup.  count_host:
 * pairs stored. */
hhg_status hhg_learn_collect(hhg_ctx* ctx, int level, const float* e0_grid_dev, int cycles, int64_t* count_host);
/* Append up to `iters` pairs from the errors of the flexible Krylov solver (CG,
 * Stokes: GCR) with the plain V-cycle on K x = f from x = 0 (f_dev FP32, nc*E, consistent
 * copies; Dirichlet values zero): the library first solves for x* (FP64 refinement to
 * 1e-10; Stokes: pressure of zero mean), then stores the pair of the error x* - x_k
 * before each preconditioner application k = 0, 1, ...  These are the errors the
 * preconditioner meets inside the solver.  count_host: pairs stored. */
hhg_status hhg_learn_collect_cg(hhg_ctx* ctx, int level, const float* f_dev, int iters, int64_t* count_host);
/* Copy stored pair `index` to the host: in_host FP32 [D][H][W][2 nc + 1] (the BF16
 * inputs), target_host FP32 [D][H][W][nc] (either nullable), nc of the stored pairs.
 * Waits. */
hhg_status hhg_learn_get_pair(hhg_ctx* ctx, int64_t index, float* in_host, float* target_host);

typedef struct {
  int steps;      /* optimiser steps */
  int batch;      /* crops per step */
  int crop;       /* crop edge in voxels (<= every pair-grid dimension) */
  double lr;      /* peak learning rate */
  uint64_t seed;  /* of the crop choices */
} hhg_learn_train_opts;

typedef struct {
  double loss_first;  /* mean loss of the first 10% of steps */
  double loss_last;   /* mean loss of the last 10% of steps */
  int64_t pairs;
  double seconds;     /* host wall time */
} hhg_learn_train_report;

/* Train on the stored pairs: each step takes `batch` random crops (pair and origin from
 * the seed), runs the forward and backward passes and one Adam step.  Waits. */
hhg_status hhg_learn_train(hhg_ctx* ctx, const hhg_learn_train_opts* opts, hhg_learn_train_report* report);
/* One preconditioner application z = a z0 + b c for the FP32 residual r_dev (nc*E)
 * (use_net = 0: z = MG(r), unscaled); alpha_host receives b / a.  Waits. */
hhg_status hhg_learn_precondition(hhg_ctx* ctx, int level, int use_net, const void* r_dev, void* z_dev,
                                  double* alpha_host);

typedef struct {
  int64_t applications;  /* preconditioner applications with the network */
  int64_t fallbacks;     /* of which fell back to the V-cycle (b = 0) */
  double alpha_mean, alpha_min, alpha_max;  /* of the weight b / a */
  double gain_mean;      /* reduction (energy norm^2; Stokes: residual norm^2) added by c,
                            relative to that of the best multiple of the multigrid step */
} hhg_learn_stats_report;

/* Statistics since the last reset (reset != 0 clears them after reading). */
hhg_status hhg_learn_stats(hhg_ctx* ctx, hhg_learn_stats_report* report, int reset);

/* End-to-end apply with host buffers: copies x_host (3*E values of type dt,
 * library layout; pinned memory gives full copy bandwidth) to a library-owned
 * device buffer, applies A (as hhg_apply) and copies the result to y_host, then
 * waits for the stream (bounded wait). */
hhg_status hhg_apply_host(hhg_ctx* ctx, int level, hhg_dtype dt, const void* x_host, void* y_host);

/* Kernel timing.  enable != 0 starts (and resets) recording CUDA events around the
 * parts of every operator sweep: the macro-interior launches (one per macro; they
 * alternate between the context stream and a side stream, so consecutive launches
 * overlap) and the skeleton kernels (on a second side stream, concurrent with the
 * interior).  ms_host[2] and launches_host[2] (nullable) receive the accumulated span
 * of each part (first start to last end, device time) and its launch count since the
 * last call; span / launches is the interior launches' effective duration.  Waits for
 * the stream. */
hhg_status hhg_profile(hhg_ctx* ctx, int enable, double* ms_host, int64_t* launches_host);

/* Kernel of the macro-interior sweeps of the scaled-stencil variants (results equal up to
 * rounding).  The point kernels take one thread per point for FP64 and, for FP32, one thread
 * per pair of neighbouring points of a lattice row in packed two-lane FP32 arithmetic, both
 * reading the stencil neighbours straight from global memory; they run either as one launch
 * per macro (the macro's stencil a kernel parameter) or as one launch over all macros (each
 * block copies its macro's stencil to shared memory), which suits meshes of many small
 * macros.  kernel: 0 (default) the point kernels, all macros in one launch when the mesh has
 * several macros and one macro's launch would fill fewer than two waves of the GPU, else one
 * launch per macro; 1 a block per 30 x 4 x 4 box of lattice points that stages the box plus
 * its one-point halo in shared memory (asynchronous copies) and reads every neighbour from
 * there; 2 the point kernels, one launch per macro; 3 the point kernels, all macros in one
 * launch.  The Stokes sweeps follow the same choice of launch shape; the colour passes of the
 * hybrid Gauss-Seidel smoother always run as one launch over all macros.  Errors: ARG for
 * another value. */
hhg_status hhg_set_interior_kernel(hhg_ctx* ctx, int kernel);

/* FP32 FMA issue-rate probe, a measurement aid with no counterpart in the paper: the
 * ALU roofline denominator of the FP32 stencil kernels.  Launches, on the context's
 * stream, one kernel of (SMs x 8) blocks of 256 threads, each thread running 8
 * independent chains of `iterations` FMAs (packed = 0: fma.rn.f32, 8 FMAs per step;
 * packed = 1: the two-lane fma.rn.f32x2, 16 FMAs per step).  out_dev: one device float
 * (written only under a condition that never holds).  flops_host receives the flops of
 * the launch (FMA = 2), sm_count_host (nullable) the device's SM count.  The caller
 * times the launch (CUDA events on the same stream).  Errors: ARG for a null pointer,
 * iterations < 1 or packed outside {0, 1}. */
hhg_status hhg_fp32_fma_probe(hhg_ctx* ctx, int packed, int64_t iterations, float* out_dev, double* flops_host,
                              int* sm_count_host);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
